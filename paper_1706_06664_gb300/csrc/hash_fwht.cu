// Structured SRP hashing (ACE_W_HADAMARD detectors; §2.2, the Fast-JL family): every block of
// dp projections of a point is the Walsh-Hadamard transform of the point with random signs,
// y = H D_b x, computed in O(dp log dp) additions by one warp per point.
//
// Layout: lane l holds coordinates e * 32 + l (e < E = dp / 32), so the loads of a row are
// coalesced, the five butterfly stages on the low index bits are shuffles across lanes and the
// rest are between a lane's own registers, and after the transform the ballot of slot e over
// the lanes is exactly the 32-bit sign word of columns b dp + 32 e .. + 31.
//
// Exactness: each output is a sum of dp terms +-x_i formed by a tree of m = log2(dp) rounded
// additions, so |y^ - y| <= gamma_m sum|x_i| (Higham, Accuracy and Stability of Numerical
// Algorithms, §4.2: any summation tree of height m), and the binary64 definition (Eq. 1 with
// this W: index-order sum of x_i w_i) is within gamma64_d sum|x_i| of y.  An output with
// |y^| > cband sum|x_i| + babs (upper bounds of both, with sum|x_i| rounded upwards) has the
// sign of the definition; the others are evaluated by the definition itself (exact_bit, binary64,
// index order) from the stored +-1 W.
#include <algorithm>

#include "fwht_plan.h"
#include "guard.cuh"

namespace ace {
namespace {

// Ids of 32 consecutive points are gathered in shared memory and stored per table with one
// point per lane (coalesced) when L * 32 ids fit kIdBufBytes; otherwise each point's ids are
// stored as it is finished.
constexpr int kIdBufBytes = 4096;

template <bool BF16, typename IdT, int E>
__global__ void __launch_bounds__(256) hash_fwht_kernel(const __grid_constant__ FwhtArgs a) {
  __shared__ uint32_t words[8][kFwhtMaxWords];
  __shared__ __align__(16) unsigned char idbuf[8][kIdBufBytes];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int d = a.d, dp = a.dp, K = a.K, L = a.L, KL = a.KL, nblk = a.nblk, mode = a.mode;
  const long long n = a.n, ld = a.ld;
  const float cband = a.cband, babs = a.babs;
  uint32_t* const wrow = words[wib];
  IdT* const ibuf = reinterpret_cast<IdT*>(idbuf[wib]);  // [L][32]
  const bool gather = static_cast<long long>(L) * 32 * static_cast<long long>(sizeof(IdT)) <= kIdBufBytes &&
                      (mode & kStoreIds) && !(mode & kStoreProj);
  const int nwords = nblk * E;
  unsigned long long nre = 0;
  // each warp takes groups of 32 consecutive points
  const long long ngroups = (n + 31) / 32;
  const long long nwarps = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
  for (long long g = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + wib; g < ngroups; g += nwarps) {
    const long long i0 = g * 32;
    const int np = static_cast<int>(min(32LL, n - i0));
    // For short rows (E <= 8) each point's loads are issued for the next point while it is
    // transformed; for long rows the registers are better spent on resident warps.
    constexpr bool kPrefetch = E <= 8;
    float xn[E];
    if constexpr (kPrefetch) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int t = e * 32 + lane;
        xn[e] = t < d ? load_x<BF16>(a.X, i0 * d + t) : 0.f;
      }
    }
    for (int p = 0; p < np; ++p) {
      const long long i = i0 + p;
      float x[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int t = e * 32 + lane;
        if constexpr (kPrefetch) {
          x[e] = xn[e];
          if (p + 1 < np) xn[e] = t < d ? load_x<BF16>(a.X, (i + 1) * d + t) : 0.f;
        } else {
          x[e] = t < d ? load_x<BF16>(a.X, i * d + t) : 0.f;
        }
      }
      float sa = 0.f, q = 0.f;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        sa = __fadd_ru(sa, fabsf(x[e]));
        q = fmaf(x[e], x[e], q);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        sa = __fadd_ru(sa, __shfl_xor_sync(0xFFFFFFFFu, sa, off));
        q += __shfl_xor_sync(0xFFFFFFFFu, q, off);
      }
      if (lane == 0 && !isfinite(q) && !(mode & kStoreProj)) atomicAdd(&a.st->nonfinite, 1ull);
      const float B = __fmaf_ru(cband, sa, babs);  // +inf or NaN for a non-finite row: all exact
      for (int b = 0; b < nblk; ++b) {
        float v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const uint32_t sw = __ldg(a.dsign + b * E + e);
          v[e] = ((sw >> lane) & 1u) ? -x[e] : x[e];
        }
        // butterflies on the lane bits (coordinates differing in bit 0..4 of t = 32 e + lane)
#pragma unroll
        for (int h = 1; h < 32; h <<= 1) {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const float o = __shfl_xor_sync(0xFFFFFFFFu, v[e], h);
            v[e] = (lane & h) ? __fsub_rn(o, v[e]) : __fadd_rn(v[e], o);
          }
        }
        // butterflies on the slot bits (bit 5.. of t)
#pragma unroll
        for (int h = 1; h < E; h <<= 1) {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            if ((e & h) == 0) {
              const float lo = v[e], hi = v[e + h];
              v[e] = __fadd_rn(lo, hi);
              v[e + h] = __fsub_rn(lo, hi);
            }
          }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int col = b * dp + e * 32 + lane;
          bool bit = v[e] > 0.f;
          if (!(fabsf(v[e]) > B) && col < KL && !(mode & kStoreProj)) {  // inside the bound (or NaN)
            bit = exact_bit<BF16>(a.X, i, d, a.Wt, col);
            ++nre;
          }
          if ((mode & kStoreProj) && col < KL) a.proj[i * static_cast<long long>(KL) + col] = v[e];
          const uint32_t wv = __ballot_sync(0xFFFFFFFFu, bit);
          if (lane == 0) wrow[b * E + e] = wv;
        }
      }
      __syncwarp();
      if (!(mode & kStoreProj)) {
        for (int j = lane; j < L; j += 32) {
          const uint32_t id = extract_bits(wrow, nwords, j * K, K);
          if (gather) ibuf[j * 32 + p] = static_cast<IdT>(id);
          else if (mode & kStoreIds) reinterpret_cast<IdT*>(a.ids)[static_cast<size_t>(j) * ld + i] = static_cast<IdT>(id);
          if (mode & kStoreIdsRowMajor) a.ids_rm[i * L + j] = id;
        }
      }
      __syncwarp();  // the words are rewritten for the next point
    }
    if (gather) {  // table j of the group's points: one point per lane
      for (int j = 0; j < L; ++j)
        if (lane < np) reinterpret_cast<IdT*>(a.ids)[static_cast<size_t>(j) * ld + i0 + lane] = ibuf[j * 32 + lane];
      __syncwarp();
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nre += __shfl_xor_sync(0xFFFFFFFFu, nre, off);
  if (lane == 0 && nre) atomicAdd(&a.st->rechecks, nre);
}

}  // namespace

cudaError_t launch_hash_fwht(const FwhtArgs& a, int num_sms, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int E = a.dp / 32;
  if (a.dp < 32 || a.dp > kFwhtMaxDp || (a.dp & (a.dp - 1)) || a.nblk * E > kFwhtMaxWords)
    return cudaErrorInvalidValue;
  const long long want = ((a.n + 31) / 32 + 7) / 8;  // groups of 32 points, 8 warps per block
  const unsigned grid = static_cast<unsigned>(std::min<long long>(want, static_cast<long long>(num_sms) * 8));
  auto go = [&](auto kern) -> cudaError_t {
    kern<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
  };
  const bool b16 = a.x_bf16 != 0, id16 = a.K <= 16;
#define ACE_FWHT_CASE(EV)                                                                          \
  case EV:                                                                                         \
    if (b16) return id16 ? go(hash_fwht_kernel<true, uint16_t, EV>) : go(hash_fwht_kernel<true, uint32_t, EV>); \
    return id16 ? go(hash_fwht_kernel<false, uint16_t, EV>) : go(hash_fwht_kernel<false, uint32_t, EV>);
  switch (E) {
    ACE_FWHT_CASE(1)
    ACE_FWHT_CASE(2)
    ACE_FWHT_CASE(4)
    ACE_FWHT_CASE(8)
    ACE_FWHT_CASE(16)
    ACE_FWHT_CASE(32)
    default:
      return cudaErrorInvalidValue;
  }
#undef ACE_FWHT_CASE
}

}  // namespace ace
