// BC7 (BPTC, UNORM) block decode on the CUDA cores: the paper's storage
// format for F_uv and the F3D slices (Sec. 3.4; supplement S2).
//
// A 16-byte block is a 128-bit little-endian bit string, fields LSB first:
// mode (m zeros then a one), partition, rotation, index selector, endpoint
// codes channel-major (R, G, B, then A) and within a channel subset-major,
// endpoint 0 then 1; p-bits (one per endpoint or one per subset, appended as
// the codes' new low bit); primary indices (texel order, anchors one bit
// shorter); secondary indices (modes 4, 5).  An n-bit endpoint expands to 8
// bits by bit replication; a texel is ((64 - w) e0 + w e1 + 32) >> 6 per
// channel; rotation 1..3 swaps A with R, G, B.  Byte 0 == 0 (reserved)
// decodes to (0, 0, 0, 0).
//
// The interpolation weights of the 2-, 3- and 4-bit indices are the nearest
// integers to 64 i / (2^b - 1) (never a tie: 128 i is even, (2k + 1)(2^b - 1)
// odd), computed here instead of tabulated.
#pragma once
#include <cstdint>

namespace ndgi {

// Partition shapes: bit p of a two-subset mask is texel p's subset; a
// three-subset word holds texel p's subset at bits 2p..2p+1.
__device__ const uint16_t kBc7Part2[64] = {
    0xCCCC, 0x8888, 0xEEEE, 0xECC8, 0xC880, 0xFEEC, 0xFEC8, 0xEC80, 0xC800, 0xFFEC, 0xFE80, 0xE800, 0xFFE8,
    0xFF00, 0xFFF0, 0xF000, 0xF710, 0x008E, 0x7100, 0x08CE, 0x008C, 0x7310, 0x3100, 0x8CCE, 0x088C, 0x3110,
    0x6666, 0x366C, 0x17E8, 0x0FF0, 0x718E, 0x399C, 0xAAAA, 0xF0F0, 0x5A5A, 0x33CC, 0x3C3C, 0x55AA, 0x9696,
    0xA55A, 0x73CE, 0x13C8, 0x324C, 0x3BDC, 0x6996, 0xC33C, 0x9966, 0x0660, 0x0272, 0x04E4, 0x4E40, 0x2720,
    0xC936, 0x936C, 0x39C6, 0x639C, 0x9336, 0x9CC6, 0x817E, 0xE718, 0xCCF0, 0x0FCC, 0x7744, 0xEE22};

__host__ __device__ constexpr uint32_t bc7_subsets3(const char (&s)[17]) {
  uint32_t w = 0;
  for (int i = 0; i < 16; ++i) w |= (uint32_t)(s[i] - '0') << (2 * i);
  return w;
}

__device__ const uint32_t kBc7Part3[64] = {
    bc7_subsets3("0011001102212222"), bc7_subsets3("0001001122112221"), bc7_subsets3("0000200122112211"),
    bc7_subsets3("0222002200110111"), bc7_subsets3("0000000011221122"), bc7_subsets3("0011001100220022"),
    bc7_subsets3("0022002211111111"), bc7_subsets3("0011001122112211"), bc7_subsets3("0000000011112222"),
    bc7_subsets3("0000111111112222"), bc7_subsets3("0000111122222222"), bc7_subsets3("0012001200120012"),
    bc7_subsets3("0112011201120112"), bc7_subsets3("0122012201220122"), bc7_subsets3("0011011211221222"),
    bc7_subsets3("0011200122002220"), bc7_subsets3("0001001101121122"), bc7_subsets3("0111001120012200"),
    bc7_subsets3("0000112211221122"), bc7_subsets3("0022002200221111"), bc7_subsets3("0111011102220222"),
    bc7_subsets3("0001000122212221"), bc7_subsets3("0000001101220122"), bc7_subsets3("0000110022102210"),
    bc7_subsets3("0122012200110000"), bc7_subsets3("0012001211222222"), bc7_subsets3("0110122112210110"),
    bc7_subsets3("0000011012211221"), bc7_subsets3("0022110211020022"), bc7_subsets3("0110011020022222"),
    bc7_subsets3("0011012201220011"), bc7_subsets3("0000200022112221"), bc7_subsets3("0000000211221222"),
    bc7_subsets3("0222002200120011"), bc7_subsets3("0011001200220222"), bc7_subsets3("0120012001200120"),
    bc7_subsets3("0000111122220000"), bc7_subsets3("0120120120120120"), bc7_subsets3("0120201212010120"),
    bc7_subsets3("0011220011220011"), bc7_subsets3("0011112222000011"), bc7_subsets3("0101010122222222"),
    bc7_subsets3("0000000021212121"), bc7_subsets3("0022112200221122"), bc7_subsets3("0022001100220011"),
    bc7_subsets3("0220122102201221"), bc7_subsets3("0101222222220101"), bc7_subsets3("0000212121212121"),
    bc7_subsets3("0101010101012222"), bc7_subsets3("0222011102220111"), bc7_subsets3("0002111200021112"),
    bc7_subsets3("0000211221122112"), bc7_subsets3("0222011101110222"), bc7_subsets3("0002111211120002"),
    bc7_subsets3("0110011001102222"), bc7_subsets3("0000000021122112"), bc7_subsets3("0110011022222222"),
    bc7_subsets3("0022001100110022"), bc7_subsets3("0022112211220022"), bc7_subsets3("0000000000002112"),
    bc7_subsets3("0002000100020001"), bc7_subsets3("0222122202221222"), bc7_subsets3("0101222222222222"),
    bc7_subsets3("0111201122012220")};

// Anchor texels per partition: byte 0 the second subset's of the two-subset
// shape, bytes 1 and 2 the second and third subsets' of the three-subset shape.
#define NDGI_BC7_ANCHORS(a2, a3, b3) ((uint32_t)(a2) | ((uint32_t)(a3) << 8) | ((uint32_t)(b3) << 16))
__device__ const uint32_t kBc7Anchors[64] = {
    NDGI_BC7_ANCHORS(15, 3, 15),  NDGI_BC7_ANCHORS(15, 3, 8),   NDGI_BC7_ANCHORS(15, 15, 8),
    NDGI_BC7_ANCHORS(15, 15, 3),  NDGI_BC7_ANCHORS(15, 8, 15),  NDGI_BC7_ANCHORS(15, 3, 15),
    NDGI_BC7_ANCHORS(15, 15, 3),  NDGI_BC7_ANCHORS(15, 15, 8),  NDGI_BC7_ANCHORS(15, 8, 15),
    NDGI_BC7_ANCHORS(15, 8, 15),  NDGI_BC7_ANCHORS(15, 6, 15),  NDGI_BC7_ANCHORS(15, 6, 15),
    NDGI_BC7_ANCHORS(15, 6, 15),  NDGI_BC7_ANCHORS(15, 5, 15),  NDGI_BC7_ANCHORS(15, 3, 15),
    NDGI_BC7_ANCHORS(15, 3, 8),   NDGI_BC7_ANCHORS(15, 3, 15),  NDGI_BC7_ANCHORS(2, 3, 8),
    NDGI_BC7_ANCHORS(8, 8, 15),   NDGI_BC7_ANCHORS(2, 15, 3),   NDGI_BC7_ANCHORS(2, 3, 15),
    NDGI_BC7_ANCHORS(8, 3, 8),    NDGI_BC7_ANCHORS(8, 6, 15),   NDGI_BC7_ANCHORS(15, 10, 8),
    NDGI_BC7_ANCHORS(2, 5, 3),    NDGI_BC7_ANCHORS(8, 8, 15),   NDGI_BC7_ANCHORS(2, 8, 6),
    NDGI_BC7_ANCHORS(2, 6, 10),   NDGI_BC7_ANCHORS(8, 8, 15),   NDGI_BC7_ANCHORS(8, 5, 15),
    NDGI_BC7_ANCHORS(2, 15, 10),  NDGI_BC7_ANCHORS(2, 15, 8),   NDGI_BC7_ANCHORS(15, 8, 15),
    NDGI_BC7_ANCHORS(15, 15, 3),  NDGI_BC7_ANCHORS(6, 3, 15),   NDGI_BC7_ANCHORS(8, 5, 10),
    NDGI_BC7_ANCHORS(2, 6, 10),   NDGI_BC7_ANCHORS(8, 10, 8),   NDGI_BC7_ANCHORS(15, 8, 9),
    NDGI_BC7_ANCHORS(15, 15, 10), NDGI_BC7_ANCHORS(2, 15, 6),   NDGI_BC7_ANCHORS(8, 3, 15),
    NDGI_BC7_ANCHORS(2, 15, 8),   NDGI_BC7_ANCHORS(2, 5, 15),   NDGI_BC7_ANCHORS(2, 15, 3),
    NDGI_BC7_ANCHORS(15, 15, 6),  NDGI_BC7_ANCHORS(15, 15, 6),  NDGI_BC7_ANCHORS(6, 15, 8),
    NDGI_BC7_ANCHORS(6, 3, 15),   NDGI_BC7_ANCHORS(2, 15, 3),   NDGI_BC7_ANCHORS(6, 5, 15),
    NDGI_BC7_ANCHORS(8, 5, 15),   NDGI_BC7_ANCHORS(15, 5, 15),  NDGI_BC7_ANCHORS(15, 8, 15),
    NDGI_BC7_ANCHORS(2, 5, 15),   NDGI_BC7_ANCHORS(2, 10, 15),  NDGI_BC7_ANCHORS(15, 5, 15),
    NDGI_BC7_ANCHORS(15, 10, 15), NDGI_BC7_ANCHORS(15, 8, 15),  NDGI_BC7_ANCHORS(15, 13, 15),
    NDGI_BC7_ANCHORS(15, 15, 3),  NDGI_BC7_ANCHORS(2, 12, 15),  NDGI_BC7_ANCHORS(2, 3, 15),
    NDGI_BC7_ANCHORS(15, 3, 8)};
#undef NDGI_BC7_ANCHORS

// Field widths of a mode:
// subsets, partition bits, rotation bits, selector bits, colour bits, alpha bits,
// p-bit per endpoint, p-bit per subset, index bits, secondary index bits.
struct Bc7Mode {
  int ns, pb, rb, isb, cb, ab, epb, spb, ib, ib2;
};

__device__ __forceinline__ Bc7Mode bc7_mode(int m) {
  switch (m) {
    case 0: return {3, 4, 0, 0, 4, 0, 1, 0, 3, 0};
    case 1: return {2, 6, 0, 0, 6, 0, 0, 1, 3, 0};
    case 2: return {3, 6, 0, 0, 5, 0, 0, 0, 2, 0};
    case 3: return {2, 6, 0, 0, 7, 0, 1, 0, 2, 0};
    case 4: return {1, 0, 2, 1, 5, 6, 0, 0, 2, 3};
    case 5: return {1, 0, 2, 0, 7, 8, 0, 0, 2, 2};
    case 6: return {1, 0, 0, 0, 7, 7, 1, 0, 4, 0};
    default: return {2, 6, 0, 0, 5, 5, 1, 0, 2, 0};
  }
}

// n bits (n <= 32) of the 128-bit block at bit pos.
__device__ __forceinline__ uint32_t bc7_bits(uint64_t lo, uint64_t hi, int pos, int n) {
  uint64_t v;
  if (pos >= 64) v = hi >> (pos - 64);
  else if (pos == 0) v = lo;
  else v = (lo >> pos) | (hi << (64 - pos));
  return (uint32_t)v & ((n >= 32) ? 0xffffffffu : ((1u << n) - 1u));
}

__device__ __forceinline__ int bc7_expand(int c, int n) { return n >= 8 ? c : (c << (8 - n)) | (c >> (2 * n - 8)); }

// Mode-6 endpoint of 8-bit channel values q[4]: the p-bit is their majority
// parity (0 on a 2-2 tie), each channel the nearest value of that parity (the
// lower on a tie).  Returns p; E[c] = 2 max(0, (q[c] - p) >> 1) + p.
__host__ __device__ __forceinline__ int bc7_mode6_endpoint(const int (&q)[4], int (&E)[4]) {
  const int odd = (q[0] & 1) + (q[1] & 1) + (q[2] & 1) + (q[3] & 1);
  const int p = odd > 2 ? 1 : 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int h = (q[c] - p) >> 1;
    E[c] = 2 * (h < 0 ? 0 : h) + p;
  }
  return p;
}

// Interpolation weight of index i of a b-bit index (b = 2, 3, 4).
__device__ __forceinline__ int bc7_weight(int i, int b) {
  const float r = b == 2 ? 64.0f / 3.0f : b == 3 ? 64.0f / 7.0f : 64.0f / 15.0f;
  return __float2int_rn((float)i * r);
}

__device__ __forceinline__ int bc7_subset(int ns, int part, int p) {
  if (ns == 2) return (__ldg(&kBc7Part2[part]) >> p) & 1;
  if (ns == 3) return (__ldg(&kBc7Part3[part]) >> (2 * p)) & 3;
  return 0;
}

// Parsed header of a block: field positions and widths.
struct Bc7Head {
  uint64_t lo, hi;
  Bc7Mode M;
  int mode, part, rot, isb;
  int ep_pos;     // first endpoint code
  int pb_pos;     // first p-bit
  int idx_pos;    // first primary index
  int anchor1, anchor2;   // anchors of subsets 1 and 2 (16: none)
};

__device__ __forceinline__ bool bc7_head(uint4 b, Bc7Head& h) {
  h.lo = (uint64_t)b.x | ((uint64_t)b.y << 32);
  h.hi = (uint64_t)b.z | ((uint64_t)b.w << 32);
  const uint32_t m0 = b.x & 0xffu;
  if (m0 == 0) return false;
  h.mode = __ffs(m0) - 1;
  h.M = bc7_mode(h.mode);
  int pos = h.mode + 1;
  h.part = (int)bc7_bits(h.lo, h.hi, pos, h.M.pb);
  pos += h.M.pb;
  h.rot = (int)bc7_bits(h.lo, h.hi, pos, h.M.rb);
  pos += h.M.rb;
  h.isb = (int)bc7_bits(h.lo, h.hi, pos, h.M.isb);
  pos += h.M.isb;
  h.ep_pos = pos;
  h.pb_pos = pos + 3 * 2 * h.M.ns * h.M.cb + 2 * h.M.ns * h.M.ab;
  h.idx_pos = h.pb_pos + (h.M.epb ? 2 * h.M.ns : h.M.spb ? h.M.ns : 0);
  h.anchor1 = h.anchor2 = 16;
  if (h.M.ns > 1) {
    const uint32_t a = __ldg(&kBc7Anchors[h.part]);
    if (h.M.ns == 2) {
      h.anchor1 = (int)(a & 0xffu);
    } else {
      h.anchor1 = (int)((a >> 8) & 0xffu);
      h.anchor2 = (int)((a >> 16) & 0xffu);
    }
  }
  return true;
}

// Expanded 8-bit endpoint e of subset s, RGBA packed (R in the low byte).
__device__ __forceinline__ uint32_t bc7_endpoint(const Bc7Head& h, int s, int e) {
  const Bc7Mode& M = h.M;
  int p = 0, pn = 0;
  if (M.epb) {
    p = (int)bc7_bits(h.lo, h.hi, h.pb_pos + 2 * s + e, 1);
    pn = 1;
  } else if (M.spb) {
    p = (int)bc7_bits(h.lo, h.hi, h.pb_pos + s, 1);
    pn = 1;
  }
  uint32_t out = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int code = (int)bc7_bits(h.lo, h.hi, h.ep_pos + (c * M.ns * 2 + s * 2 + e) * M.cb, M.cb);
    out |= (uint32_t)bc7_expand(pn ? (code << 1) | p : code, M.cb + pn) << (8 * c);
  }
  int a = 255;
  if (M.ab) {
    const int code = (int)bc7_bits(h.lo, h.hi, h.ep_pos + 3 * M.ns * 2 * M.cb + (s * 2 + e) * M.ab, M.ab);
    a = bc7_expand(pn ? (code << 1) | p : code, M.ab + pn);
  }
  return out | ((uint32_t)a << 24);
}

// Interpolates packed endpoints: colour with weight wc, alpha with weight wa; applies the rotation.
__device__ __forceinline__ uint32_t bc7_mix(uint32_t e0, uint32_t e1, int wc, int wa, int rot) {
  uint32_t v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int w = c < 3 ? wc : wa;
    const int a = (int)((e0 >> (8 * c)) & 0xffu), b = (int)((e1 >> (8 * c)) & 0xffu);
    v[c] = (uint32_t)(((64 - w) * a + w * b + 32) >> 6);
  }
  if (rot) {
    const uint32_t t = v[3];
    v[3] = v[rot - 1];
    v[rot - 1] = t;
  }
  return v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24);
}

// Index bits of texel p: position of its primary index and width.
__device__ __forceinline__ void bc7_index1(const Bc7Head& h, int p, int& pos, int& n) {
  const int before = (p > 0) + (h.anchor1 < p) + (h.anchor2 < p);
  const bool anchor = p == 0 || p == h.anchor1 || p == h.anchor2;
  pos = h.idx_pos + p * h.M.ib - before;
  n = h.M.ib - (anchor ? 1 : 0);
}

// RGBA8 (R in the low byte) of texel p (= 4 row + col) of a block.
__device__ __forceinline__ uint32_t bc7_texel(uint4 b, int p) {
  Bc7Head h;
  if (!bc7_head(b, h)) return 0u;
  const int s = bc7_subset(h.M.ns, h.part, p);
  const uint32_t e0 = bc7_endpoint(h, s, 0), e1 = bc7_endpoint(h, s, 1);
  int pos, n;
  bc7_index1(h, p, pos, n);
  const int i1 = (int)bc7_bits(h.lo, h.hi, pos, n);
  int wc = bc7_weight(i1, h.M.ib), wa = wc;
  if (h.M.ib2) {
    const int pos2 = h.idx_pos + 16 * h.M.ib - 1 + p * h.M.ib2 - (p > 0);
    const int i2 = (int)bc7_bits(h.lo, h.hi, pos2, h.M.ib2 - (p == 0));
    const int w2 = bc7_weight(i2, h.M.ib2);
    if (h.isb) wc = w2;
    else wa = w2;
  }
  return bc7_mix(e0, e1, wc, wa, h.rot);
}

// All sixteen texels of a block (RGBA8, texel p at out[p]).
__device__ __forceinline__ void bc7_block(uint4 b, uint32_t (&out)[16]) {
  Bc7Head h;
  if (!bc7_head(b, h)) {
#pragma unroll
    for (int p = 0; p < 16; ++p) out[p] = 0u;
    return;
  }
  uint32_t e[3][2];
#pragma unroll
  for (int s = 0; s < 3; ++s)
    if (s < h.M.ns) {
      e[s][0] = bc7_endpoint(h, s, 0);
      e[s][1] = bc7_endpoint(h, s, 1);
    } else {
      e[s][0] = e[s][1] = 0u;
    }
  int pos = h.idx_pos, pos2 = h.idx_pos + 16 * h.M.ib - 1;
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    const bool anchor = p == 0 || p == h.anchor1 || p == h.anchor2;
    const int n = h.M.ib - (anchor ? 1 : 0);
    const int i1 = (int)bc7_bits(h.lo, h.hi, pos, n);
    pos += n;
    int wc = bc7_weight(i1, h.M.ib), wa = wc;
    if (h.M.ib2) {
      const int n2 = h.M.ib2 - (p == 0);
      const int w2 = bc7_weight((int)bc7_bits(h.lo, h.hi, pos2, n2), h.M.ib2);
      pos2 += n2;
      if (h.isb) wc = w2;
      else wa = w2;
    }
    const int s = bc7_subset(h.M.ns, h.part, p);
    const uint32_t a = s == 0 ? e[0][0] : s == 1 ? e[1][0] : e[2][0];
    const uint32_t c = s == 0 ? e[0][1] : s == 1 ? e[1][1] : e[2][1];
    out[p] = bc7_mix(a, c, wc, wa, h.rot);
  }
}

}  // namespace ndgi
