// Resolution of the (point, table) pairs that the tensor-core hash kernel deferred: their
// K bits recomputed exactly, binary32 first, then the Dot2 filter, then the binary64
// definition of Eq. 1 for what neither can decide.
#include "guard.cuh"
#include "tc_plan.h"

namespace ace {
namespace {

// Resolves the deferred (point, table) pairs, one pair per lane: the lane reads the point's
// coordinates once and recomputes the table's K columns as K binary32 FMA chains in index
// order, each with the binary32 sum of the magnitudes of its partial sums (the running error
// bound), and decides each column with the smaller of two rigorous bounds on its distance
// from the binary64 definition: the SIMT engine's a priori bound (gamma_d sum|x_i w_i| +
// d 2^-150, folded into cB32[c] ||x||_up + babs32) and the chain's running bound (u / (1 - u)
// times that sum, plus the binary64 sum's own error), which is several times tighter where
// the sum crosses zero -- exactly the deferred columns.  A column inside both goes to the
// Dot2 filter, and only what Dot2 cannot decide is evaluated in binary64, index order (the
// definition).  GB300 issues binary64 FMAs at a small fraction of the binary32 rate, so the
// filters keep that path to exact ties.  With one pair per lane a warp keeps 32 pairs in
// flight, so the pass is bound by issue rather than by the latency of dependent rounds.
// KM: the largest K of the instantiation (16 for 16-bit ids, 24 otherwise).
template <bool BF16, typename IdT, int KM>
__global__ void __launch_bounds__(256) recheck_kernel(const __grid_constant__ TcArgs a, int nseg) {
  const int d = a.d, K = a.K, L = a.L, mode = a.mode, dp = a.dp;
  const long long ld = a.ld;
  const int seg = blockIdx.y;
  if (seg >= nseg) return;
  const unsigned long long cnt = a.defer_counts[seg];
  const unsigned long long* const list = a.defer + a.seg_cap * static_cast<unsigned long long>(seg);
  IdT* const ids = reinterpret_cast<IdT*>(a.ids);
  const float xfac32 = a.xfac32, xabs32 = a.xabs32, babs32 = a.babs32;
  const float runc = a.runc, run64 = a.run64, runabs = a.runabs;
  unsigned long long nre = 0;
  for (unsigned long long e = static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < cnt;
       e += static_cast<unsigned long long>(gridDim.x) * blockDim.x) {
    const unsigned long long w = list[e];
    const long long i = static_cast<long long>(w >> 24);
    const int j = static_cast<int>(w & 0xFFFFFFull);
    const float* const wc = a.Wp + static_cast<size_t>(j) * K * dp;  // column j K + k at wc + k dp
    float s[KM], run[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) s[k] = run[k] = 0.f;
    float q = 0.f;
    const long long xb = i * d;
    // index order; Wp rows are zero-padded to dp (a multiple of 4): the padding adds exact zeros
    for (int t = 0; t < dp; t += 4) {
      float xv[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) xv[m] = t + m < d ? load_x<BF16>(a.X, xb + t + m) : 0.f;
#pragma unroll
      for (int m = 0; m < 4; ++m) q = fmaf(xv[m], xv[m], q);
#pragma unroll
      for (int k = 0; k < KM; ++k) {
        if (k < K) {
          const float4 w4 = __ldg(reinterpret_cast<const float4*>(wc + static_cast<size_t>(k) * dp + t));
          s[k] = fmaf(xv[0], w4.x, s[k]);
          run[k] = __fadd_rn(run[k], fabsf(s[k]));
          s[k] = fmaf(xv[1], w4.y, s[k]);
          run[k] = __fadd_rn(run[k], fabsf(s[k]));
          s[k] = fmaf(xv[2], w4.z, s[k]);
          run[k] = __fadd_rn(run[k], fabsf(s[k]));
          s[k] = fmaf(xv[3], w4.w, s[k]);
          run[k] = __fadd_rn(run[k], fabsf(s[k]));
        }
      }
    }
    const float xu = norm_upper(q, xfac32, xabs32);
    uint32_t id = 0u;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      if (k < K) {
        const int col = j * K + k;
        const float cb = __ldg(a.cB32 + col);
        const float brun = __fmaf_ru(runc, run[k], __fmaf_ru(__fmul_ru(run64, cb), xu, runabs));
        bool bit;
        if (fabsf(s[k]) > fminf(fmaf(cb, xu, babs32), brun)) {
          bit = s[k] > 0.f;
        } else {
          const int sg = dot2_sign<BF16>(a.X, i, d, a.Wp + static_cast<size_t>(col) * dp, 1, a.dot2c, a.dot2abs);
          bit = sg != 0 ? sg > 0 : exact_bit<BF16>(a.X, i, d, a.Wt, col);
        }
        id |= (bit ? 1u : 0u) << k;
      }
    }
    if (mode & kTagDeferred) {  // the insert pass skips this table: count it here
      ids[static_cast<size_t>(j) * ld + i] = static_cast<IdT>(id | 0x8000u);
      atomicAdd(a.counts + (static_cast<size_t>(j) << K) + id, 1u);
    } else if (mode & kStoreIds) {
      ids[static_cast<size_t>(j) * ld + i] = static_cast<IdT>(id);
    }
    if (mode & kStoreIdsRowMajor) a.ids_rm[i * L + j] = id;
    nre += static_cast<unsigned long long>(K);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nre += __shfl_xor_sync(0xFFFFFFFFu, nre, off);
  if ((threadIdx.x & 31) == 0 && nre) atomicAdd(&a.st->rechecks, nre);
}

}  // namespace

cudaError_t launch_recheck(const TcArgs& a, int num_sms, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int nseg = static_cast<int>(min(static_cast<long long>(num_sms), a.ntiles));  // one segment per CTA
  // one pair per lane: a few blocks per segment (a segment holds a few hundred pairs at the
  // KDD shape); a block loops when its segment holds more
  auto go = [&](auto kern) -> cudaError_t {
    const dim3 grid(4, static_cast<unsigned>(nseg));
    kern<<<grid, 256, 0, s>>>(a, nseg);
    return cudaGetLastError();
  };
  const bool id16 = a.K <= 16;
  if (a.x_bf16) return id16 ? go(recheck_kernel<true, uint16_t, 16>) : go(recheck_kernel<true, uint32_t, 24>);
  return id16 ? go(recheck_kernel<false, uint16_t, 16>) : go(recheck_kernel<false, uint32_t, 24>);
}

}  // namespace ace
