// Device code of the query phase, shared by the score kernels (count_kernels.cu) and the
// persistent batched kernel (hash_simt.cu): exact 128-bit folds of S1 = sum c and S2 = sum c^2,
// the correctly rounded derivation of mu, sigma and the threshold (§5.3), one block of the
// gather of Algorithm 1's query phase, and one block of scores and flags.
#pragma once

#include "ace_internal.h"

namespace ace {
namespace {

__device__ __forceinline__ void add128(unsigned long long& lo, unsigned long long& hi, unsigned long long l2,
                                       unsigned long long h2) {
  const unsigned long long s = lo + l2;
  hi += h2 + (s < lo ? 1ull : 0ull);
  lo = s;
}

// Exact: the sum modulo 2^128 is independent of the order of the atomics.
__device__ __forceinline__ void atomic_add128(unsigned long long* p, unsigned long long lo, unsigned long long hi) {
  if (lo) {
    const unsigned long long old = atomicAdd(p, lo);
    if (old + lo < old) hi += 1ull;
  }
  if (hi) atomicAdd(p + 1, hi);
}

// Block-wide sum of (s1 as 64-bit, s2 as 128-bit); thread 0 adds it to the globals.
__device__ void block_fold(unsigned long long s1, unsigned long long s2lo, unsigned long long s2hi,
                           unsigned long long* S1, unsigned long long* S2) {
  __shared__ unsigned long long sh[3][32];
  unsigned long long s1hi = 0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long a = __shfl_down_sync(0xFFFFFFFFu, s1, off);
    const unsigned long long b = __shfl_down_sync(0xFFFFFFFFu, s1hi, off);
    const unsigned long long c = __shfl_down_sync(0xFFFFFFFFu, s2lo, off);
    const unsigned long long d = __shfl_down_sync(0xFFFFFFFFu, s2hi, off);
    add128(s1, s1hi, a, b);
    add128(s2lo, s2hi, c, d);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ unsigned long long sh1hi[32];
  if (lane == 0) {
    sh[0][w] = s1;
    sh1hi[w] = s1hi;
    sh[1][w] = s2lo;
    sh[2][w] = s2hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, ah = 0, b = 0, bh = 0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) {
      add128(a, ah, sh[0][i], sh1hi[i]);
      add128(b, bh, sh[1][i], sh[2][i]);
    }
    atomic_add128(S1, a, ah);
    atomic_add128(S2, b, bh);
  }
}

// Correctly rounded (nearest-even) conversion of a 128-bit unsigned integer to binary64.
__device__ double u128_to_f64(unsigned long long lo, unsigned long long hi) {
  if (hi == 0) return __ull2double_rn(lo);
  const int s = __clzll(static_cast<long long>(hi));
  unsigned long long top = s == 0 ? hi : ((hi << s) | (lo >> (64 - s)));
  const unsigned long long rest = lo << s;
  top |= rest != 0 ? 1ull : 0ull;  // sticky bit, below the rounding position of a 64-bit value
  const double scale = __longlong_as_double(static_cast<long long>(1023 + 64 - s) << 52);
  return __dmul_rn(__ull2double_rn(top), scale);
}

// mu, sigma and t from the folded N, S1, S2 (called once, by the last block to fold).
__device__ void finish_stats(DevStats* st, int L, double alpha) {
  volatile DevStats* v = st;
  const unsigned long long N = v->n_scored;
  const unsigned long long s1lo = v->S1[0], s1hi = v->S1[1], s2lo = v->S2[0], s2hi = v->S2[1];
  // N * S2 as 128 bits, with overflow detection
  const unsigned long long plo = N * s2lo;
  const unsigned long long pmid = __umul64hi(N, s2lo);
  const unsigned long long hlo = N * s2hi;
  const bool ovf = __umul64hi(N, s2hi) != 0 || pmid + hlo < pmid || s1hi != 0 || N == 0;
  const unsigned long long phi = pmid + hlo;
  // S1^2 (S1 < 2^64 whenever N*S2 < 2^128, by Cauchy-Schwarz)
  const unsigned long long qlo = s1lo * s1lo, qhi = __umul64hi(s1lo, s1lo);
  const unsigned long long vlo = plo - qlo;
  const unsigned long long vhi = phi - qhi - (plo < qlo ? 1ull : 0ull);
  double mu, sigma, t;
  if (ovf) {
    if (N != 0) atomicOr(&st->status, static_cast<unsigned>(ACE_STATUS_SUM_OVERFLOW));
    mu = sigma = t = __longlong_as_double(0x7ff8000000000000LL);
  } else {
    const double NL = __dmul_rn(__ull2double_rn(N), static_cast<double>(L));
    mu = __ddiv_rn(u128_to_f64(s1lo, s1hi), NL);
    sigma = __ddiv_rn(__dsqrt_rn(u128_to_f64(vlo, vhi)), NL);
    t = __dsub_rn(mu, __dmul_rn(alpha, sigma));
  }
  st->mu = mu;
  st->sigma = sigma;
  st->threshold = t;
}

// Block `blk` of `nblocks` of one detector's query phase.  Returns true in thread 0 of the block
// that derived mu, sigma and the threshold (the last to fold).  NC: the counts may be read
// through the read-only cache (they do not change during the kernel); otherwise they are read
// from L2 (the persistent batched kernel writes them earlier in the same launch).
template <typename IdT, bool NC = true>
__device__ __forceinline__ bool score_block(const IdT* __restrict__ ids, long long ld, long long n, int K, int L,
                                            double alpha, const uint32_t* __restrict__ counts,
                                            uint32_t* __restrict__ sums, DevStats* st, long long blk,
                                            long long nblocks) {
  const long long i = blk * blockDim.x + threadIdx.x;
  unsigned long long c = 0;
  if (i < n) {
    const IdT* col = ids + i;
    const uint32_t kmask = (1u << K) - 1u;  // drops the deferred-table tag (16-bit ids, K <= 15)
#pragma unroll 10
    for (int j = 0; j < L; ++j) {
      const uint32_t id = col[static_cast<size_t>(j) * ld] & kmask;
      c += NC ? __ldg(counts + (static_cast<size_t>(j) << K) + id) : __ldcg(counts + (static_cast<size_t>(j) << K) + id);
    }
    if (c > 0xFFFFFFFFull) atomicOr(&st->status, static_cast<unsigned>(ACE_STATUS_SUM_OVERFLOW));
    sums[i] = static_cast<uint32_t>(c);
  }
  block_fold(c, c * c, __umul64hi(c, c), st->S1, st->S2);
  if (threadIdx.x == 0) {
    if (blk == 0) atomicAdd(&st->n_scored, static_cast<unsigned long long>(n));
    // the last block to fold (after every other block's sums are visible) derives mu, sigma, t
    __threadfence();
    const unsigned int ticket = atomicAdd(&st->done, 1u);
    if (ticket == nblocks - 1) {
      __threadfence();
      finish_stats(st, L, alpha);
      st->done = 0u;
      return true;
    }
  }
  return false;
}

// One block of a detector's scores and flags: score = RN(c / L) by integer arithmetic;
// flag = score < t, compared on bit patterns (scores are non-negative, so their order is that
// of their bits; a threshold that is not positive, NaN included, flags nothing).
// (threshold and sums are read from L2: the persistent batched kernel writes them earlier in the
// same launch)
__device__ __forceinline__ void flags_block(const ScoreJob& j, long long blk) {
  const long long i = blk * blockDim.x + threadIdx.x;
  if (i >= j.n) return;
  const long long tb = __double_as_longlong(__ldcg(&j.st->threshold));
  const bool tpos = tb > 0 && tb <= 0x7ff0000000000000LL;
  const unsigned long long sb = rn_quotient_bits(__ldcg(j.sums + i), j.div);
  if (j.scores) j.scores[i] = __longlong_as_double(static_cast<long long>(sb));
  if (j.flags) j.flags[i] = (tpos && static_cast<long long>(sb) < tb) ? 1 : 0;
}

}  // namespace
}  // namespace ace
