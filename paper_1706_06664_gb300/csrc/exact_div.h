// The score of §3.2, c / L, as the correctly rounded (nearest) binary64 quotient of two
// integers, computed with integer arithmetic only (GB300 issues binary64 instructions at a
// small fraction of its integer rate).  Host and device share this header, so a host test
// can check it against an exact rational reference.
//
// Method.  Write L = 2^z Lo with Lo odd; then c / L = (c / Lo) 2^-z and rounding commutes with
// the power of two (the quotients here are far from the subnormal range).  Normalise c to
// cn = c 2^sh in [2^31, 2^32).  With M = floor(2^96 / Lo), the 128-bit product A = cn M
// satisfies X - 2^32 < A <= X for X = 2^96 cn / Lo.  With Lo < 2^16 (the detector's K L <=
// 65536 gives L <= 65536), A >= 2^127 / Lo - 2^32 has its leading bit p >= 111.  A
// rounding midpoint m is an odd multiple of 2^(p-53), and X - m = (cn 2^96 - m Lo) / Lo whose
// numerator is an even multiple of 2^(p-53) minus an odd one, so |X - m| >= 2^(p-53) / Lo >=
// 2^(p-69) >= 2^42.  A is therefore on the same side of every midpoint as X (and no tie
// occurs), so rounding A to 53 bits by its first dropped bit gives RN(X).  When Lo = 1 the
// quotient is exact.
#pragma once

#include <cassert>
#include <cstdint>

#if defined(__CUDACC__)
#define ACE_HD __host__ __device__ __forceinline__
#else
#define ACE_HD inline
#endif

namespace ace {

struct DivConst {
  uint64_t m_lo;  // M = floor(2^96 / Lo) = m_hi 2^64 + m_lo (unused when Lo = 1)
  uint32_t m_hi;
  int z;          // L = 2^z Lo
  int pow2;       // 1 when Lo = 1
};

// Host: the constants of divisor L.  Precondition: 1 <= L <= 65536 (so the odd part Lo of L
// is below 2^16, which the rounding argument above needs).
inline DivConst make_div_const(uint32_t L) {
  assert(L >= 1u && L <= 65536u);
  DivConst k{};
  uint32_t lo = L;
  while ((lo & 1u) == 0u) {
    lo >>= 1;
    ++k.z;
  }
  k.pow2 = lo == 1u;
  if (!k.pow2) {
    const unsigned __int128 M = (static_cast<unsigned __int128>(1) << 96) / lo;
    k.m_hi = static_cast<uint32_t>(M >> 64);
    k.m_lo = static_cast<uint64_t>(M);
  }
  return k;
}

ACE_HD int ace_clz32(uint32_t v) {
#if defined(__CUDA_ARCH__)
  return __clz(static_cast<int>(v));
#else
  return __builtin_clz(v);
#endif
}
ACE_HD int ace_clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return __clzll(static_cast<long long>(v));
#else
  return __builtin_clzll(v);
#endif
}
ACE_HD uint64_t ace_mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return static_cast<uint64_t>((static_cast<unsigned __int128>(a) * b) >> 64);
#endif
}

// Bits of the binary64 value RN(c / L) for the divisor whose constants are k.
ACE_HD uint64_t rn_quotient_bits(uint32_t c, const DivConst& k) {
  if (c == 0u) return 0ull;
  const int sh = ace_clz32(c);
  const uint64_t cn = static_cast<uint64_t>(c) << sh;  // leading bit at 31
  constexpr uint64_t kFrac = (1ull << 52) - 1ull;
  if (k.pow2) {
    const int e = 31 - sh - k.z;
    return (static_cast<uint64_t>(e + 1023) << 52) | ((cn << 21) & kFrac);
  }
  const uint64_t lo = cn * k.m_lo;
  const uint64_t hi = ace_mulhi64(cn, k.m_lo) + cn * static_cast<uint64_t>(k.m_hi);  // A = hi 2^64 + lo
  const int s = ace_clz64(hi);                                                       // 1 <= s <= 16
  const uint64_t w = (hi << s) | (lo >> (64 - s));                                 // leading bit at 63
  uint64_t mant = (w >> 11) + ((w >> 10) & 1ull);
  int e = (127 - s) - 96 - sh - k.z;
  if (mant >> 53) {
    mant >>= 1;
    ++e;
  }
  return (static_cast<uint64_t>(e + 1023) << 52) | (mant & kFrac);
}

}  // namespace ace
