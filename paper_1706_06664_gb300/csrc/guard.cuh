// Device helpers shared by the hash kernels: input loads, the Dot2 filter and the exact
// binary64 recheck.
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

// Binary64 sum of x_i w_i in index order (the definition's sum, Eq. 1); Wt is [KL][d].
template <bool BF16>
__device__ __forceinline__ double exact_sum(const void* X, long long i, int d, const float* Wt, int col) {
  const long long base = i * static_cast<long long>(d);
  const float* w = Wt + static_cast<size_t>(col) * static_cast<size_t>(d);
  double s = 0.0;
#pragma unroll 8
  for (int k = 0; k < d; ++k)  // unrolled so that the loads run ahead; the order of the sum is kept
    s = fma(static_cast<double>(load_x<BF16>(X, base + k)), static_cast<double>(__ldg(w + k)), s);
  return s;
}

// Exact SRP bit of point i on column col: binary64, index order.
template <bool BF16>
__device__ __noinline__ bool exact_bit(const void* X, long long i, int d, const float* Wt, int col) {
  return exact_sum<BF16>(X, i, d, Wt, col) > 0.0;
}

// The same bit with a binary64 term added to the sum at the end (the privacy noise of §4.5):
// [RN(s + add) > 0], which has the sign of s + add.
template <bool BF16>
__device__ __noinline__ bool exact_bit_add(const void* X, long long i, int d, const float* Wt, int col, double add) {
  return __dadd_rn(exact_sum<BF16>(X, i, d, Wt, col), add) > 0.0;
}

// Dot2 (Ogita, Rump & Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6),
// 2005): binary32 error-free transformations (TwoProduct by FMA, Knuth's TwoSum) carry the
// sum of x_i w_i in about twice the working precision; without underflow the result res
// satisfies |res - x.w| <= u |x.w| + gamma_d^2 sum|x_i w_i|.  Returns res; a = the computed
// sum of |x_i w_i|.  Every operation is an explicitly rounded intrinsic, so no contraction
// into an FMA can break the transformations.  w is read with stride ws.
template <bool BF16>
__device__ __forceinline__ float dot2_sum(const void* X, long long i, int d, const float* w, long long ws, float& a) {
  const long long base = i * static_cast<long long>(d);
  float p = 0.f, e = 0.f;
  a = 0.f;
#pragma unroll 4
  for (int k = 0; k < d; ++k) {
    const float x = load_x<BF16>(X, base + k);
    const float y = __ldg(w + k * ws);
    const float h = __fmul_rn(x, y);
    const float r = __fmaf_rn(x, y, -h);  // h + r = x y exactly (TwoProduct)
    const float p1 = __fadd_rn(p, h);
    const float z = __fsub_rn(p1, p);
    const float q = __fadd_rn(__fsub_rn(p, __fsub_rn(p1, z)), __fsub_rn(h, z));  // p1 + q = p + h (TwoSum)
    p = p1;
    e = __fadd_rn(e, __fadd_rn(q, r));
    a = __fadd_rn(a, fabsf(h));
  }
  return __fadd_rn(p, e);
}

// Sign of the exact dot product x.w by Dot2.  When |res| exceeds gamma_d^2 sum|x_i w_i| plus
// the binary64 sum's own error gamma64_d sum|x_i w_i|, the exact value and the binary64
// definition both have the sign of res and are non-zero (the relative term u |x.w| cannot
// change a sign).  c2 covers those terms together with the rounding of the computed sum of
// |x_i w_i|; cabs covers underflow.  Returns +1 or -1 when decided, 0 when only binary64 can
// tell (exact ties, NaN, overflow).
template <bool BF16>
__device__ __noinline__ int dot2_sign(const void* X, long long i, int d, const float* w, long long ws, float c2,
                                      float cabs) {
  float a;
  const float res = dot2_sum<BF16>(X, i, d, w, ws, a);
  const float T = __fmaf_ru(c2, a, cabs);
  if (fabsf(res) > T) return res > 0.f ? 1 : -1;  // false for NaN, and for any res when T = inf
  return 0;
}

// Sign of x.w + add (the privacy noise of §4.5: add is the binary32 eta, whose binary64 value
// differs by at most 2^-24 |add|).  The relative term of Dot2's bound now matters (u |x.w| <=
// u |res| (1 + 2u)), and the final addition rounds once more (2^-24 |res + add|): the bound
// gains 2^-23 (|res| + |add| + |res + add|), twice those terms.
template <bool BF16>
__device__ __noinline__ int dot2_sign_add(const void* X, long long i, int d, const float* w, long long ws, float c2,
                                          float cabs, float add) {
  float a;
  const float res = dot2_sum<BF16>(X, i, d, w, ws, a);
  const float v = __fadd_rn(res, add);
  float T = __fmaf_ru(c2, a, cabs);
  T = __fmaf_ru(1.1920928955078125e-07f, __fadd_ru(__fadd_ru(fabsf(res), fabsf(add)), fabsf(v)), T);
  if (fabsf(v) > T) return v > 0.f ? 1 : -1;
  return 0;
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
