// The fits' counter-based sample stream (shared by fit.cu and hybrid_fit.cu).
#pragma once
#include <cstdint>

namespace ndgi {

// ---------------------------------------------------------------------------
// Counter-based sample stream: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Sample i of step `step`: texel (ix, iy) and t = (z2 >> 40) 2^-24, a 24-bit
// fraction in [0, 1) (exact in FP32).
__device__ __forceinline__ void draw_sample(uint64_t seed, int64_t step, int64_t i, int lm_w, int lm_h, int& ix,
                                            int& iy, float& t) {
  const uint64_t g = 0x9E3779B97F4A7C15ull;
  const uint64_t ctr = ((uint64_t)step << 32) + (uint64_t)i;
  const uint64_t base = seed + 2ull * ctr * g;
  const uint64_t z1 = splitmix64(base);
  const uint64_t z2 = splitmix64(base + g);
  ix = (int)((uint32_t)z1 % (uint32_t)lm_w);
  iy = (int)((uint32_t)(z1 >> 32) % (uint32_t)lm_h);
  t = (float)(uint32_t)(z2 >> 40) * 0x1p-24f;
}

}  // namespace ndgi
