// Exact resolution of structured-projection outputs (ACE_W_HADAMARD): the whole warp of a
// point evaluates one output y_t = sum_i D_b[i] H[t][i] x_i with the row in registers (lane l
// holds coordinates 32 e + l, zero beyond d) as a binary64 sum, exact in any order when the
// row's coordinates span few enough binades.
#pragma once

#include <cstdint>

namespace ace {

// Whether every binary64 sum of +-x_t (t < dp) is exact for this row: all coordinates finite,
// and the sums' bits, from the lowest significant bit of the smallest non-zero |x_t|
// (2^(E_t - 150), or 2^(E_t - 134) for bfloat16 values, with the biased exponent E_t >= 1) to
// the top of dp 2^(E_max - 126), fit binary64's 53.  Then the sum's value does not depend on the
// order of the additions: a warp can split it.  (The warp's x registers hold the row.)
template <bool BF16, int E>
__device__ __forceinline__ bool exact_tier_applies(const float (&x)[E], int m) {
  uint32_t emax = 0u, emin = 255u;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t u = __float_as_uint(x[e]) & 0x7FFFFFFFu;
    const uint32_t ef = u >> 23;
    emax = max(emax, ef);
    if (u) emin = min(emin, max(ef, 1u));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, off));
    emin = min(emin, __shfl_xor_sync(0xFFFFFFFFu, emin, off));
  }
  if (emax >= 255u) return false;  // inf or NaN
  if (emax == 0u && emin == 255u) return true;  // a zero row
  const int lo = static_cast<int>(emin) - (BF16 ? 134 : 150);
  const int hi = static_cast<int>(emax) - 126 + m;
  return hi - lo <= 53;
}

// The sum over t of W[t][b dp + j] x_t with W[t][c] = D_b[t] H[j][t] (fm: this lane's sign bits
// of block b, bit e for t = 32 e + lane), in binary64: each lane adds its E terms, the warp
// joins the lanes' sums.  Exact when exact_tier_applies; every lane returns the same value.
template <int E>
__device__ __forceinline__ double coop_sum(const float (&x)[E], uint32_t fm, int j, int lane) {
  const uint32_t lp = static_cast<uint32_t>(__popc(static_cast<uint32_t>(j & 31) & static_cast<uint32_t>(lane))) & 1u;
  const uint32_t jh = static_cast<uint32_t>(j) >> 5;
  double s = 0.0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t neg = ((fm >> e) ^ lp ^ static_cast<uint32_t>(__popc(jh & static_cast<uint32_t>(e)))) & 1u;
    s = __dadd_rn(s, neg ? -static_cast<double>(x[e]) : static_cast<double>(x[e]));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xFFFFFFFFu, s, off));
  return s;
}

}  // namespace ace
