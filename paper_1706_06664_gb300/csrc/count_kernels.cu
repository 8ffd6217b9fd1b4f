// Query phase and score statistics.
//
//   score_gather  Algorithm 1 query phase (§3.2): c_i = sum_j A_j[H_j(q_i)] from the cached
//                 table-major ids; folds N += n, S1 += sum c, S2 += sum c^2 (exact 128-bit);
//                 its last block derives the §5.3 threshold once: mu = S1/(N L),
//                 sigma = sqrt(N S2 - S1^2)/(N L), t = mu - alpha*sigma.  Every binary64 step is
//                 an explicit correctly rounded intrinsic, so no contraction can change it.
//   flags         score = c/L (correctly rounded, integer arithmetic) and flag = score < t.
//   sum_squares   Q = sum over all counters of A^2 (the closed form of Eq. 11 summed over
//                 the inserts: mu_ins = Q / (n_ins L)).
#include <algorithm>

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

// Block `blk` of `nblocks` of one detector's query phase.
template <typename IdT>
__device__ __forceinline__ void score_block(const IdT* __restrict__ ids, long long ld, long long n, int K, int L,
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
      c += __ldg(counts + (static_cast<size_t>(j) << K) + id);
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
    }
  }
}

template <typename IdT>
__global__ void __launch_bounds__(256) score_gather_kernel(const IdT* __restrict__ ids, long long ld, long long n, int K,
                                                           int L, double alpha, const uint32_t* __restrict__ counts,
                                                           uint32_t* __restrict__ sums, DevStats* st) {
  score_block<IdT>(ids, ld, n, K, L, alpha, counts, sums, st, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ int job_of(const long long* __restrict__ start, int ndet, long long b) {
  int lo = 0, hi = ndet;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Many detectors' query phases in one launch (blocks of detector g: [start[g], start[g+1])).
template <typename IdT>
__global__ void __launch_bounds__(256) score_batched_kernel(const ScoreJob* __restrict__ jobs,
                                                            const long long* __restrict__ start, int ndet) {
  const long long total = start[ndet];
  for (long long b = blockIdx.x; b < total; b += gridDim.x) {
    const int g = job_of(start, ndet, b);
    const ScoreJob& j = jobs[g];
    score_block<IdT>(static_cast<const IdT*>(j.ids), j.ld, j.n, j.K, j.L, j.alpha, j.counts, j.sums, j.st,
                     b - start[g], start[g + 1] - start[g]);
    __syncthreads();  // block_fold's shared memory is reused by the next block
  }
}

// Many detectors' flags in one launch (same block layout as score_batched_kernel).
__global__ void __launch_bounds__(256) flags_batched_kernel(const ScoreJob* __restrict__ jobs,
                                                            const long long* __restrict__ start, int ndet) {
  const long long total = start[ndet];
  for (long long b = blockIdx.x; b < total; b += gridDim.x) {
    const int g = job_of(start, ndet, b);
    const ScoreJob& j = jobs[g];
    const long long i = (b - start[g]) * blockDim.x + threadIdx.x;
    if (i >= j.n) continue;
    const long long tb = __double_as_longlong(j.st->threshold);
    const bool tpos = tb > 0 && tb <= 0x7ff0000000000000LL;
    const unsigned long long sb = rn_quotient_bits(j.sums[i], j.div);
    if (j.scores) j.scores[i] = __longlong_as_double(static_cast<long long>(sb));
    if (j.flags) j.flags[i] = (tpos && static_cast<long long>(sb) < tb) ? 1 : 0;
  }
}

// score = RN(c / L) by integer arithmetic; flag = score < t, compared on bit patterns (scores
// are non-negative, so their order is that of their bits; a threshold that is not positive,
// NaN included, flags nothing).
__global__ void __launch_bounds__(256) flags_kernel(const uint32_t* __restrict__ sums, long long n, DivConst div,
                                                    const DevStats* __restrict__ st, double* __restrict__ scores,
                                                    uint8_t* __restrict__ flags) {
  const long long tb = __double_as_longlong(st->threshold);
  const bool tpos = tb > 0 && tb <= 0x7ff0000000000000LL;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const unsigned long long sb = rn_quotient_bits(sums[i], div);
    if (scores) scores[i] = __longlong_as_double(static_cast<long long>(sb));
    if (flags) flags[i] = (tpos && static_cast<long long>(sb) < tb) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(256) sum_squares_kernel(const uint32_t* __restrict__ counts, long long total,
                                                          DevStats* st) {
  unsigned long long lo = 0, hi = 0;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const unsigned long long c = counts[i];
    add128(lo, hi, c * c, 0ull);
  }
  // reuse the 128-bit fold: (0, Q) -> S1 slot unused
  __shared__ unsigned long long sh[2][32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long a = __shfl_down_sync(0xFFFFFFFFu, lo, off);
    const unsigned long long b = __shfl_down_sync(0xFFFFFFFFu, hi, off);
    add128(lo, hi, a, b);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][w] = lo;
    sh[1][w] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, ah = 0;
    for (int i = 0; i < static_cast<int>((blockDim.x + 31) >> 5); ++i) add128(a, ah, sh[0][i], sh[1][i]);
    atomic_add128(st->Q, a, ah);
  }
}

constexpr size_t kHistBytes = 128 * 1024;  // shared-memory histogram of one insert block

// Counting phase (Algorithm 1; §3.2) from cached table-major ids: A_j[id] += 1 for every
// point.  Block (j, part, range) owns table j, bucket slice `part` (all 2^K buckets when they
// fit in kHistBytes) and one range of points; it counts into a shared-memory histogram, then
// adds the non-zero bins to A_j with one global atomic each.  The ids are read with 16-byte
// loads over the aligned middle of the range.  Counts are exact integers, so the order of
// the additions is irrelevant.
template <typename IdT>
__global__ void __launch_bounds__(1024) insert_hist_kernel(const IdT* __restrict__ ids, long long ld, long long n,
                                                           int K, int nparts, int nranges,
                                                           uint32_t* __restrict__ counts) {
  extern __shared__ uint32_t hist[];
  const int bins = (1 << K) / nparts;
  const int j = blockIdx.x / (nparts * nranges);
  const int part = (blockIdx.x / nranges) % nparts;
  const int rr = blockIdx.x % nranges;
  const long long per = ((n + nranges - 1) / nranges + 7) & ~7LL;
  const long long i0 = min(n, rr * per);
  const long long i1 = min(n, i0 + per);
  const uint32_t lo = static_cast<uint32_t>(part) * static_cast<uint32_t>(bins);
  for (int b = threadIdx.x; b < bins; b += blockDim.x) hist[b] = 0u;
  __syncthreads();
  const IdT* col = ids + static_cast<size_t>(j) * ld;
  auto add = [&](uint32_t id) {
    const uint32_t rel = id - lo;
    if (rel < static_cast<uint32_t>(bins)) atomicAdd(&hist[rel], 1u);
  };
  constexpr int V = 16 / sizeof(IdT);  // ids per 16-byte load
  const long long mis =
      static_cast<long long>((16 - (reinterpret_cast<uintptr_t>(col + i0) & 15)) & 15) / static_cast<long long>(sizeof(IdT));
  const long long h1 = min(i1, i0 + mis);  // first 16-byte-aligned id of the range
  const long long nvec = (i1 - h1) / V;
  const long long t0 = h1 + nvec * V;  // scalar tail [t0, i1)
  for (long long i = i0 + threadIdx.x; i < h1; i += blockDim.x) add(col[i]);
  const uint4* vp = reinterpret_cast<const uint4*>(col + h1);
  for (long long v = threadIdx.x; v < nvec; v += blockDim.x) {
    const uint4 u = vp[v];
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if constexpr (sizeof(IdT) == 2) {
        add(w[k] & 0xFFFFu);
        add(w[k] >> 16);
      } else {
        add(w[k]);
      }
    }
  }
  for (long long i = t0 + threadIdx.x; i < i1; i += blockDim.x) add(col[i]);
  __syncthreads();
  uint32_t* dst = counts + (static_cast<size_t>(j) << K) + lo;
  for (int b = threadIdx.x; b < bins; b += blockDim.x) {
    const uint32_t v = hist[b];
    if (v) atomicAdd(dst + b, v);
  }
}

// Same counting for wide tables (K > 16): warp-merged global atomics.
template <typename IdT>
__global__ void __launch_bounds__(256) insert_direct_kernel(const IdT* __restrict__ ids, long long ld, long long n,
                                                            int K, int L, uint32_t* __restrict__ counts) {
  const long long total = n * L;
  for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int j = static_cast<int>(e / n);
    const long long i = e - static_cast<long long>(j) * n;
    atomicAdd(counts + (static_cast<size_t>(j) << K) + ids[static_cast<size_t>(j) * ld + i], 1u);
  }
}

// Deletion (§3.4.1), checked before it is applied: a bucket whose count is below the batch's
// histogram means a point of the batch was never inserted.
__global__ void __launch_bounds__(256) delete_check_kernel(const uint32_t* __restrict__ hist,
                                                           const uint32_t* __restrict__ counts, long long total,
                                                           unsigned int* __restrict__ flag) {
  bool bad = false;
  for (long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += static_cast<long long>(gridDim.x) * blockDim.x)
    bad |= hist[t] > counts[t];
  if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

__global__ void __launch_bounds__(256) delete_apply_kernel(const uint32_t* __restrict__ hist, uint32_t* __restrict__ counts,
                                                           long long total) {
  for (long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += static_cast<long long>(gridDim.x) * blockDim.x)
    counts[t] -= hist[t];
}

// Sliding-window eviction (§3.4.1 deletion of the oldest points): for the m oldest points of
// the ring [L][cap] (starting at slot `start`, wrapping), A_j[id] -= 1 for every table j.
template <typename IdT>
__global__ void __launch_bounds__(256) window_evict_kernel(const IdT* __restrict__ ring, long long cap, long long start,
                                                           long long m, int K, int L, uint32_t* __restrict__ counts) {
  const long long total = m * L;
  for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int j = static_cast<int>(e / m);
    long long p = start + (e - static_cast<long long>(j) * m);
    if (p >= cap) p -= cap;
    // (16-bit ids of the tensor-core insert path may carry the deferred-table tag, bit 15 > K)
    const uint32_t id = static_cast<uint32_t>(ring[static_cast<size_t>(j) * cap + p]) & ((1u << K) - 1u);
    atomicSub(counts + (static_cast<size_t>(j) << K) + id, 1u);
  }
}

}  // namespace

cudaError_t launch_window_evict(const void* ring, int ids16, long long cap, long long start, long long m, int K, int L,
                                uint32_t* counts, int num_sms, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((m * L + 255) / 256, static_cast<long long>(num_sms) * 8);
  if (ids16)
    window_evict_kernel<uint16_t><<<static_cast<unsigned>(blocks), 256, 0, s>>>(static_cast<const uint16_t*>(ring), cap,
                                                                                start, m, K, L, counts);
  else
    window_evict_kernel<uint32_t><<<static_cast<unsigned>(blocks), 256, 0, s>>>(static_cast<const uint32_t*>(ring), cap,
                                                                                start, m, K, L, counts);
  return cudaGetLastError();
}

cudaError_t launch_score_batched(const ScoreJob* jobs_dev, const long long* start_dev, int ndet, bool id16, int num_sms,
                                 cudaStream_t s) {
  const unsigned grid = static_cast<unsigned>(num_sms * 8);
  if (id16) score_batched_kernel<uint16_t><<<grid, 256, 0, s>>>(jobs_dev, start_dev, ndet);
  else score_batched_kernel<uint32_t><<<grid, 256, 0, s>>>(jobs_dev, start_dev, ndet);
  return cudaGetLastError();
}

cudaError_t launch_flags_batched(const ScoreJob* jobs_dev, const long long* start_dev, int ndet, int num_sms,
                                 cudaStream_t s) {
  flags_batched_kernel<<<static_cast<unsigned>(num_sms * 8), 256, 0, s>>>(jobs_dev, start_dev, ndet);
  return cudaGetLastError();
}

cudaError_t launch_delete_check(const uint32_t* hist, const uint32_t* counts, long long total, unsigned int* flag,
                                int num_sms, cudaStream_t s) {
  const long long blocks = std::min<long long>((total + 255) / 256, static_cast<long long>(num_sms) * 8);
  delete_check_kernel<<<static_cast<unsigned>(std::max<long long>(1, blocks)), 256, 0, s>>>(hist, counts, total, flag);
  return cudaGetLastError();
}

cudaError_t launch_delete_apply(const uint32_t* hist, uint32_t* counts, long long total, int num_sms, cudaStream_t s) {
  const long long blocks = std::min<long long>((total + 255) / 256, static_cast<long long>(num_sms) * 8);
  delete_apply_kernel<<<static_cast<unsigned>(std::max<long long>(1, blocks)), 256, 0, s>>>(hist, counts, total);
  return cudaGetLastError();
}

cudaError_t launch_insert_from_ids(const void* ids, int ids16, long long ld, long long n, int K, int L,
                                   uint32_t* counts, int num_sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (K <= 16) {
    // the fewest bucket slices whose histogram fits in kHistBytes of shared memory
    int nparts = 1;
    while ((static_cast<size_t>(1) << K) / nparts * sizeof(uint32_t) > kHistBytes) nparts *= 2;
    const int bins = (1 << K) / nparts;
    const size_t smem = static_cast<size_t>(bins) * sizeof(uint32_t);
    auto go = [&](auto kern, const auto* typed) -> cudaError_t {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 1024, smem);
      if (e != cudaSuccess) return e;
      // one wave: split each (table, slice) into point ranges until the SMs are covered
      const long long units = static_cast<long long>(L) * nparts;
      const long long want = static_cast<long long>(num_sms) * max(1, per_sm);
      const long long nranges = max(1LL, min(want / units, (n + 4095) / 4096));
      kern<<<static_cast<unsigned>(units * nranges), 1024, smem, s>>>(typed, ld, n, K, nparts,
                                                                       static_cast<int>(nranges), counts);
      return cudaGetLastError();
    };
    if (ids16) return go(insert_hist_kernel<uint16_t>, static_cast<const uint16_t*>(ids));
    return go(insert_hist_kernel<uint32_t>, static_cast<const uint32_t*>(ids));
  }
  const unsigned blocks = static_cast<unsigned>(num_sms * 8);
  if (ids16)
    insert_direct_kernel<uint16_t><<<blocks, 256, 0, s>>>(static_cast<const uint16_t*>(ids), ld, n, K, L, counts);
  else
    insert_direct_kernel<uint32_t><<<blocks, 256, 0, s>>>(static_cast<const uint32_t*>(ids), ld, n, K, L, counts);
  return cudaGetLastError();
}

cudaError_t launch_score_gather(const void* ids, int ids16, long long ld, long long n, int K, int L, double alpha,
                                const uint32_t* counts, uint32_t* sums, DevStats* st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = (n + 255) / 256;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (ids16)
    score_gather_kernel<uint16_t><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
        static_cast<const uint16_t*>(ids), ld, n, K, L, alpha, counts, sums, st);
  else
    score_gather_kernel<uint32_t><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
        static_cast<const uint32_t*>(ids), ld, n, K, L, alpha, counts, sums, st);
  return cudaGetLastError();
}

cudaError_t launch_flags(const uint32_t* sums, long long n, const DivConst& div, const DevStats* st, double* scores,
                         uint8_t* flags, cudaStream_t s) {
  if (n <= 0 || (!scores && !flags)) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  flags_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(sums, n, div, st, scores, flags);
  return cudaGetLastError();
}

cudaError_t launch_sum_squares(const uint32_t* counts, long long total, DevStats* st, cudaStream_t s) {
  long long blocks = (total + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 152 * 8) blocks = 152 * 8;
  sum_squares_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(counts, total, st);
  return cudaGetLastError();
}

}  // namespace ace
