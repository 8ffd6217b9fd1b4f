// Projection matrix of Algorithm 1's hash initialisation step (§3.2): K*L Gaussian vectors,
// w_i ~ N(0,1) (§2.1), drawn on the host from a 64-bit seed.
//
// Generator (published definitions): SplitMix64 of Steele, Lea and Flood (OOPSLA 2014),
// read in counter mode — draw t of seed s is the SplitMix64 finaliser applied to
// s + (t+1) * 0x9E3779B97F4A7C15 — and the Box-Muller transform (1958) on consecutive
// pairs of draws.  Pair p gives u1 = ((draw_{2p} >> 11) + 1) * 2^-53 in (0, 1] and
// u2 = (draw_{2p+1} >> 11) * 2^-53 in [0, 1); with r = sqrt(-2 ln u1) and a = 2 pi u2,
// flat element 2p is r cos a and flat element 2p+1 is r sin a, each rounded to binary32.
// The flat index of W[i][c] is i*K*L + c.
//
// Built with -ffp-contract=off and -fno-builtin so that each binary64 step is one
// correctly rounded operation and libm's cos/sin/log/sqrt are called as written.
// With ACE_W_BF16 each binary32 value is then rounded to bfloat16 (round_projection_bf16).
#include <cmath>
#include <cstdint>
#include <cstring>

#include "ace_internal.h"
#include "fwht_plan.h"

namespace ace {

namespace {

inline uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

inline uint64_t draw(uint64_t seed, uint64_t t) { return mix64(seed + (t + 1u) * 0x9E3779B97F4A7C15ull); }

}  // namespace

// bfloat16 bit pattern of a finite binary32 value, round to nearest even.
inline uint16_t to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return static_cast<uint16_t>((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

void round_projection_bf16(float* W, uint64_t total) {
  for (uint64_t i = 0; i < total; ++i) {
    const uint32_t u = static_cast<uint32_t>(to_bf16(W[i])) << 16;
    std::memcpy(&W[i], &u, 4);
  }
}

void generate_projection_hadamard(int d, int K, int L, uint64_t seed, float* W, uint32_t* dsign) {
  const int KL = K * L, dp = fwht_order(d), nblk = (KL + dp - 1) / dp;
  for (int b = 0; b < nblk; ++b)
    for (int w = 0; w < dp / 32; ++w) {
      uint32_t word = 0;
      for (int t = 0; t < 32; ++t)
        if (draw(seed, static_cast<uint64_t>(b) * dp + 32u * w + t) & 1u) word |= 1u << t;
      dsign[b * (dp / 32) + w] = word;
    }
  for (int i = 0; i < d; ++i)
    for (int c = 0; c < KL; ++c) {
      const int b = c / dp, j = c % dp;
      const bool neg_d = (dsign[b * (dp / 32) + i / 32] >> (i % 32)) & 1u;
      const bool neg_h = __builtin_popcount(static_cast<unsigned>(i & j)) & 1;
      W[static_cast<size_t>(i) * KL + c] = (neg_d != neg_h) ? -1.0f : 1.0f;
    }
}

void generate_projection_counter(int d, int K, int L, uint64_t seed, float* W) {
  const uint64_t total = static_cast<uint64_t>(d) * static_cast<uint64_t>(K) * static_cast<uint64_t>(L);
  for (uint64_t f = 0; f < total; ++f) W[f] = counter_w(seed, f);
}

void generate_projection(int d, int K, int L, uint64_t seed, float* W) {
  const uint64_t total = static_cast<uint64_t>(d) * static_cast<uint64_t>(K) * static_cast<uint64_t>(L);
  const double two_pi = 2.0 * 3.14159265358979323846;
  for (uint64_t p = 0; 2 * p < total; ++p) {
    const uint64_t a = draw(seed, 2 * p);
    const uint64_t b = draw(seed, 2 * p + 1);
    const double u1 = static_cast<double>((a >> 11) + 1u) * 0x1.0p-53;
    const double u2 = static_cast<double>(b >> 11) * 0x1.0p-53;
    const double lg = std::log(u1);
    const double r = std::sqrt(-2.0 * lg);
    const double angle = two_pi * u2;
    const double c = std::cos(angle);
    W[2 * p] = static_cast<float>(r * c);
    if (2 * p + 1 < total) {
      const double s = std::sin(angle);
      W[2 * p + 1] = static_cast<float>(r * s);
    }
  }
}

}  // namespace ace
