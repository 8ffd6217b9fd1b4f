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
#include "score_block.cuh"
#include "launch_cache.h"

namespace ace {
namespace {

template <typename IdT>
__global__ void __launch_bounds__(256) score_gather_kernel(const IdT* __restrict__ ids, long long ld, long long n, int K,
                                                           int L, double alpha, const uint32_t* __restrict__ counts,
                                                           uint32_t* __restrict__ sums, DevStats* st) {
  score_block<IdT>(ids, ld, n, K, L, alpha, counts, sums, st, blockIdx.x, gridDim.x);
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
      cudaError_t e = smem_limit(kern, static_cast<int>(smem));
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      e = blocks_per_sm(&per_sm, kern, 1024, smem);
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
