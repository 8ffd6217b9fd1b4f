// Device helpers shared by the hash kernels: input loads and the exact binary64 recheck.
//
// The SRP bit of Eq. 1 is defined here as [s > 0] with s the binary64 sum, in index order,
// of the products (double)x_i * (double)w_i.  A binary32 x binary32 (or bfloat16 x binary32)
// product has at most 48 significant bits, so it is exact in binary64 and fma(x, w, s)
// rounds exactly like s + x*w.  A fast path that lands inside its error bound calls
// exact_bit(), which evaluates that definition literally.
#pragma once

#include "ace_internal.h"

namespace ace {

template <bool BF16>
__device__ __forceinline__ float load_x(const void* X, long long idx) {
  if constexpr (BF16) {
    const unsigned short h = __ldg(reinterpret_cast<const unsigned short*>(X) + idx);
    return __uint_as_float(static_cast<unsigned>(h) << 16);
  } else {
    return __ldg(reinterpret_cast<const float*>(X) + idx);
  }
}

// Exact SRP bit of point i on column col: binary64, index order, Wt is [KL][d].
template <bool BF16>
__device__ __noinline__ bool exact_bit(const void* X, long long i, int d, const float* Wt, int col) {
  const long long base = i * static_cast<long long>(d);
  const float* w = Wt + static_cast<size_t>(col) * static_cast<size_t>(d);
  double s = 0.0;
  for (int k = 0; k < d; ++k)
    s = fma(static_cast<double>(load_x<BF16>(X, base + k)), static_cast<double>(__ldg(w + k)), s);
  return s > 0.0;
}

// K (<= 24) consecutive bits starting at bit `cb` of a row of 32-bit words.
__device__ __forceinline__ uint32_t extract_bits(const uint32_t* row, int nwords, int cb, int K) {
  const int w = cb >> 5, sh = cb & 31;
  unsigned long long v = row[w];
  if (w + 1 < nwords) v |= static_cast<unsigned long long>(row[w + 1]) << 32;
  return static_cast<uint32_t>(v >> sh) & ((1u << K) - 1u);
}

// Upper bound of ||x||_2 from the binary32 sum of squares q (any summation order):
// |q^ - q| <= gamma_d q + d 2^-150, so sqrt(q^ * xfac + xabs) rounded up covers ||x||.
// A non-finite q (NaN/Inf coordinate or overflow) gives +inf: every projection of the
// point is then recomputed in binary64.
__device__ __forceinline__ float norm_upper(float q, float xfac, float xabs) {
  if (!isfinite(q)) return __int_as_float(0x7f800000);
  return sqrtf(fmaf(q, xfac, xabs)) * 1.00000095367431640625f;  // (1 + 2^-20)
}

}  // namespace ace
